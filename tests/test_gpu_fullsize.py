"""Parity at the full workload sizes, in the configuration the benchmark times (batched; the
mixed FP32 operators + FP64 refinement, and the FP64 operators), against the oracle's
single-domain FP64 solve (dense or banded LAPACK Cholesky of the assembled system A u = f,
Sec. 2.3.3), element by element:

* decomposition and B bit-exact against the oracle's construction;
* a sampled assembled subdomain matrix against the oracle's subdomain assembly (<= 5e-12
  of its largest entry: summation order of up to ~10^3 FP64 contributions per entry);
* every right-hand side's nodal solution within a relative nodal error of 1e-8 (max over the
  non-Dirichlet dofs of |u - u*| / max |u*|) of the oracle's, for both precisions: the
  accuracy the solver targets (the FETI solution equals the single-domain one, Sec. 4).

The workloads: 1-D constant kernel (999 dofs, 4 parts, 1 RHS), 2-D constant l2 kernel
(16129 dofs, 4 x 4, 8 RHS), 2-D fractional s = 0.5, delta = 0.2 (9025 dofs, 6 x 6 with
Omega_k = empty on the interior parts, all 64 RHS) and 2-D peridynamics (130050 dofs, 8 x 8
jittered, 36 floating parts with 3 rigid modes, all 16 RHS).
Edge case: a single right-hand side of the same problem equals the batched column.
"""
import numpy as np
import pytest

import workloads as W
from oracle import assembly
from oracle.decomposition import build_decomposition
from oracle import problem as oprob

pytestmark = pytest.mark.gpu

FULL = {
    "const_1d": W.const_1d,
    "const_l2_2d": W.const_l2_2d,
    "fractional_2d": W.fractional_2d,
    "peridynamic_2d": W.peridynamic_2d,
}


@pytest.fixture(scope="module")
def ctx():
    from paper_2306_00094_gb300 import binding
    return binding.Context()


@pytest.mark.parametrize("name", list(FULL))
def test_full_size(ctx, name):
    from paper_2306_00094_gb300 import binding
    w = FULL[name]()
    nc = w.kernel.ncomp
    p = binding.Problem.from_workload(ctx, w)
    dec = build_decomposition(w.mesh, w.kernel, w.labels, w.K)
    d = p.decomposition()
    assert np.array_equal(d["nodes"], np.concatenate([s.nodes for s in dec.subs]))
    assert np.array_equal(d["B_plus"], dec.B_plus) and np.array_equal(d["B_minus"], dec.B_minus)
    assert np.array_equal(d["floating"].astype(bool), dec.floating)
    # sampled rows of one subdomain matrix
    rng = np.random.default_rng(0)
    k = int(rng.integers(dec.K))
    dofs = dec.dofs(k)
    dof_of = np.full(w.mesh.n_nodes * nc, -1, np.int32)
    dof_of[dofs] = np.arange(dofs.size, dtype=np.int32)
    Ak_ref, _ = assembly.assemble(w.mesh, w.kernel, w.kernel.scale, dof_of, dofs.size, elem_mask=dec.elem_mask, k=k)
    Ak = p.operator(k, 0)
    assert np.abs(Ak - Ak_ref).max() <= 5e-12 * np.abs(Ak_ref).max()
    del Ak, Ak_ref
    # the oracle's single-domain solution of every right-hand side
    ref = oprob.Monolithic(w.mesh, w.kernel).solve(w.rhs, w.rhs_kind)
    p.factor(3)
    for precision in (1, 0):
        p.set_options(binding.default_options(precision=precision, batched=1))
        u, st = p.solve(w.rhs, w.rhs_kind)
        err = oprob.rel_nodal_error(u, ref, w.mesh, nc)
        assert err.shape == (w.nrhs,)
        assert (err <= 1e-8).all(), (precision, err.max(), st)
        if precision == 1:
            # a single right-hand side of the same problem equals the batched column
            u1, _ = p.solve(w.rhs[:, :1], w.rhs_kind)
            assert np.abs(u1[:, 0] - u[:, 0]).max() <= 1e-9 * np.abs(u[:, 0]).max()
    p.close()
