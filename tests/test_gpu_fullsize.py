"""Parity at the full workload sizes, in the configuration the benchmark times (batched, mixed
FP32 operators + FP64 refinement), on outputs the oracle can produce one by one:

* decomposition and B bit-exact against the oracle's construction;
* a sampled assembled subdomain matrix against the oracle's subdomain assembly (<= 5e-12
  of its largest entry: summation order of up to ~10^3 FP64 contributions per entry);
* the solution satisfies sampled rows of the oracle's single-domain system: for a relative
  nodal error of 1e-8 the row residual is bounded by 1e-8 * sum_j |A_ij| |u_j| (times a
  small safety factor).
Edge cases: a ragged right-hand-side count (11) and a single right-hand side.
"""
import numpy as np
import pytest

import workloads as W
from oracle import assembly
from oracle.decomposition import build_decomposition
from oracle import problem as oprob

pytestmark = pytest.mark.gpu

FULL = {
    "const_1d": lambda: W.const_1d(),
    "const_l2_2d": lambda: W.const_l2_2d(),
    "fractional_2d": lambda: W.fractional_2d(nrhs=11),
    "peridynamic_2d": lambda: W.peridynamic_2d(nrhs=1),
}


@pytest.fixture(scope="module")
def ctx():
    from paper_2306_00094_gb300 import binding
    return binding.Context()


@pytest.mark.parametrize("name", list(FULL))
def test_full_size(ctx, name):
    from paper_2306_00094_gb300 import binding
    w = FULL[name]()
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
    dof_of = np.full(w.mesh.n_nodes * w.kernel.ncomp, -1, np.int32)
    dof_of[dofs] = np.arange(dofs.size, dtype=np.int32)
    Ak_ref, _ = assembly.assemble(w.mesh, w.kernel, w.kernel.scale, dof_of, dofs.size, elem_mask=dec.elem_mask, k=k)
    Ak = p.operator(k, 0)
    assert np.abs(Ak - Ak_ref).max() <= 5e-12 * np.abs(Ak_ref).max()
    # solve in the benchmark configuration
    p.factor(2)
    p.set_options(binding.default_options(precision=1, batched=1))
    u, st = p.solve(w.rhs, w.rhs_kind)
    nc = w.kernel.ncomp
    free = np.flatnonzero(w.mesh.node_is_dirichlet == 0)
    free_dofs = (free[:, None] * nc + np.arange(nc)[None, :]).ravel()
    rows = np.sort(rng.choice(free_dofs, size=12, replace=False))
    Arows = assembly.assemble_rows(w.mesh, w.kernel, w.kernel.scale, rows)
    F = oprob.load_vector(w.mesh, nc, w.rhs, w.rhs_kind)
    res = F[rows] - Arows @ u
    scale = np.abs(Arows) @ np.abs(u) + np.abs(F[rows])
    assert (np.abs(res) <= 1e-7 * scale).all(), (np.abs(res) / scale).max()
    # single right-hand side of the same problem equals the corresponding column
    u1, _ = p.solve(w.rhs[:, :1], w.rhs_kind)
    assert np.abs(u1[:, 0] - u[:, 0]).max() <= 1e-9 * np.abs(u[:, 0]).max()
