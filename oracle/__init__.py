"""CPU oracle for the Helmholtz MLFMA matvec.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` (and its ``--impl reference`` arm) may import,
call, link or execute anything in this package.  The GPU library never uses it,
and this package shares no code with the GPU path.

Contents
  direct  -- FP64 direct sum and gradient (plain C + OpenMP), the exact result.
  special -- Gauss-Legendre rule, spherical Bessel/Hankel, (associated) Legendre.
  tree    -- bounding cube, Morton keys, octree levels, colleague/U/V/W/X lists.
  mlfma   -- plain FP64 MLFMA with per-stage dumps (C2M, M2M, M2L, L2L, L2O, P2P).

Parity status: every function is pinned by tests/test_oracle_*.py against
library routines (numpy leggauss, scipy spherical_jn/yn, lpmv), closed forms
(h_0, single source), brute force (tiny trees, O(N^2) adjacency) and invariants
(Funk-Hecke, exact interpolation of band-limited functions, weighted adjoint,
pair-partition invariant, reciprocity).
"""
