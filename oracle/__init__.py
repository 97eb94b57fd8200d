"""FP64 CPU oracle for the nonlocal FETI solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import anything here.  The
oracle shares no code with the CUDA path (``paper_2306_00094_gb300``); both read
their inputs from ``workloads``, which holds no arithmetic of the method.

Contents, each following the paper's statement:

* ``nl_quad.c`` / ``assembly.py`` -- element-pair quadrature of the bilinear
  form (eq. bil1, eq. bilinear-multi1), single-domain and per-subdomain.
* ``decomposition.py`` -- the nonlocal subdivision (Def. nonlocalsubdivision,
  Sec. 5.1), zeta (eq. zeta), index sets I_k / G_k, B, D, B_D, Z, G.
* ``problem.py`` -- load vectors and the single-domain system A u = f - B g (Sec. 2.3.3),
  solved by Cholesky (dense or banded LAPACK).
* ``feti.py`` -- one-level FETI, Algorithm 1 with the scaled Dirichlet
  preconditioner (eq. preconditioner) and the pinning pseudo-inverse (Sec. 5.3).

Pins (tests under ``tests/test_oracle_*.py``): closed forms in 1-D and for the
l-infinity kernel in 2-D, exact kernels of the matrices, symmetry and
definiteness, partition of unity, FETI == monolithic, S S^+ S = S against an
SVD pseudo-inverse, brute-force quadrature on tiny inputs, the continuous
operator limits of the kernel constants.  Parity unpinned: the individual
matrix entries of the l2 nocaps and polar-singular rules at full size (there the
written rule plus two independent implementations is the definition).
"""
