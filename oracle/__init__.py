"""Oracle: a plain, slow, FP64 CPU statement of the hierarchical ORAS method.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; only the
test-suite, the smoke check in ``__graft_entry__`` and the CPU-baseline leg of
``bench.py`` may import or run it.  It shares no code with the CUDA path: it is
written from the paper (Gander, Jiang & Zhang, "Hierarchical Coarse Basis by
Randomised SVD: the Helmholtz Problem") and uses numpy/scipy library routines
(sparse LU, dense QR/SVD/LU) as individual steps.

Modules
-------
problem    discrete impedance Helmholtz operator and right-hand side (Eq. (1), Sec. 3.1)
hierarchy  binary strip hierarchy with overlap (Sec. 1, Sec. 3)
sketch     counter-based complex Gaussian sketch (SplitMix64 + Box-Muller)
method     O-method: ORAS sweeps, interface maps, randomised SVD, Galerkin
           coarse spaces and the hierarchical iteration (Eqs. (2)-(5), Sec. 2)
direct     O-direct: the discrete solution u* = A^{-1} b by sparse direct solve

Pins: every function here is checked by ``tests/test_oracle_*.py`` against facts the
paper or the mathematics fix (one-step exactness of the coarse-corrected iteration,
plane-wave convergence, brute-force dense solves, adjoint identities, Galerkin
orthogonality, published SplitMix64 outputs).  Parity of the randomised basis
vectors themselves beyond those pins is unpinned (they are random by design); the
tests compare subspaces and basis-independent operators instead.
"""
