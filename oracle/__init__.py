"""Plain, slow FP64 CPU oracle for the Kaehler-Dirac staggered multigrid solve.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never calls it and shares no code, tables or helpers with it; both read their
inputs from ``sw_inputs``.

What it computes follows Brower, Clark, Strelchenko and Weinberg,
"Multigrid for Staggered Lattice Fermions" (arXiv:1801.07823):

* ``lattice``   -- index maps: eta phases (Sec. II, after Eq. staggeredD), epsilon (Eq. epsilon),
                   Kaehler-Dirac blocks (Sec. II.A, Fig. BC_partition), aggregates (Table kcycle).
* ``operators`` -- staggered D (Eq. staggeredD), the block split D = B + C and
                   A = D B^-1 (Eq. defA), the Schur operator I - A_eo A_oe (Table kcycle),
                   all as explicit sparse matrices built entry by entry.
* ``krylov``    -- CG, CGNE, MR and (flexible) GCR written out step by step.
* ``mg``        -- null-vector setup, chiral doubling, block orthonormalisation,
                   Galerkin P^dag A P (Sec. III.C and IV), and the K-cycle solve.

Every function is FP64 (complex128) and uses numpy/scipy primitives (sparse
products, 4x4 inverses, vdot) as single steps, with no blocking or fusion.
Parity pins: see tests/test_oracle_*.py.  No part is "parity unpinned".
"""
